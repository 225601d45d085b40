"""Exploratory mutation sweeps over the oracle's C source (test tooling, not
collected by pytest).  Each sweep applies one kind of single-site change to
every matching site of the code after the file's definitions, compiles every
mutant on the CPU, runs the oracle's pin files against it (the driver of
test_pin_strength.py) and prints the mutants the pins did not catch.  The
named mutants of test_pin_strength.py and its lists of equivalent kinds come
from reading these survivors.

    python tests/pin_sweeps.py relational   # < <= > >= == != flipped
    python tests/pin_sweeps.py arith        # binary + and - flipped
    python tests/pin_sweeps.py literal      # integer literals moved by +-1
    python tests/pin_sweeps.py logic        # && and || flipped
    python tests/pin_sweeps.py swap         # a paired name replaced by its partner
    python tests/pin_sweeps.py delete       # a single-line statement deleted

A mutant that does not compile, crashes or runs past 60 s is reported as
such; it is not a survivor.  All sweeps together take about half an hour on
eight cores.
"""
import os
import re
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import test_pin_strength as T  # noqa: E402

SRC = open(T.SRC).read()


def _mask(s):
    """Comments and string literals blanked (positions kept)."""
    out = list(s)
    for m in re.finditer(r'/\*.*?\*/|//[^\n]*|"[^"\n]*"|#include[^\n]*|#define[^\n]*', s, flags=re.S):
        for i in range(m.start(), m.end()):
            if out[i] != "\n":
                out[i] = " "
    return "".join(out)


CODE = _mask(SRC)
START = CODE.index("double or_level_scale")


def _site(pos):
    ln = CODE.count("\n", 0, pos) + 1
    line = CODE[CODE.rfind("\n", 0, pos) + 1:CODE.find("\n", pos)].strip()
    return ln, line[:100]


def _replace(pos, old, new):
    return SRC[:pos] + new + SRC[pos + len(old):]


def relational():
    flip = {"<=": "<", ">=": ">", "<": "<=", ">": ">=", "==": "!=", "!=": "=="}
    for m in re.finditer(r"<=|>=|==|!=|(?<![<>-])<(?![<=])|(?<![<>-])>(?![>=])", CODE):
        if m.start() >= START:
            yield m.start(), _replace(m.start(), m.group(0), flip[m.group(0)]), f"{m.group(0)} -> {flip[m.group(0)]}"


def arith():
    for m in re.finditer(r"(?<=[\w\)\]]) ([+-]) (?=[\w\(])", CODE):
        if m.start() >= START:
            i = m.start(1)
            new = "-" if CODE[i] == "+" else "+"
            yield i, _replace(i, CODE[i], new), f"{CODE[i]} -> {new}"


def literal():
    for m in re.finditer(r"(?<![\w.])(\d+)(u|ull|ll)?(?![\w.])", CODE):
        if m.start() < START:
            continue
        v = int(m.group(1))
        for dv in (1, -1):
            if v + dv >= 0:
                yield m.start(), _replace(m.start(), m.group(1), str(v + dv)), f"{v} -> {v + dv}"


def logic():
    for m in re.finditer(r"&&|\|\|", CODE):
        if m.start() >= START:
            new = "||" if m.group(0) == "&&" else "&&"
            yield m.start(), _replace(m.start(), m.group(0), new), f"{m.group(0)} -> {new}"


PAIRS = [("x", "y"), ("W", "H"), ("W0", "H0"), ("dx", "dy"), ("X", "Y"), ("kl", "kr"), ("d1", "d3"), ("lc", "rc"),
         ("Lk", "Rk"), ("px", "py"), ("qx", "qy"), ("xa", "ya"), ("xb", "yb"), ("m10", "m01"), ("cx", "cy"),
         ("x0", "y0"), ("x1", "y1"), ("Wn", "Hn"), ("p00", "p01"), ("p10", "p11"), ("a", "b"), ("u", "v"), ("i", "j")]


def swap():
    partner = {}
    for a, b in PAIRS:
        partner[a], partner[b] = b, a
    for m in re.finditer(r"(?<![\w.>])([A-Za-z_]\w*)(?!\w)", CODE):
        if m.start() >= START and m.group(1) in partner:
            yield m.start(), _replace(m.start(), m.group(1), partner[m.group(1)]), f"{m.group(1)} -> {partner[m.group(1)]}"


def delete():
    decl = re.compile(r"^(int32_t|uint32_t|double|float|int64_t|uint8_t|uint16_t|size_t|or_\w+|const|int8_t|"
                      r"uint64_t|volatile|int)\b")
    pos = 0
    for line in SRC.split("\n"):
        st = line.strip()
        if (pos >= START and st.endswith(";") and "{" not in st and "}" not in st and not decl.match(st)
                and not st.startswith(("//", "*", "/*", "typedef", "static const", "return"))):
            at = pos + len(line) - len(line.lstrip())
            yield at, _replace(at, st, ";"), "statement deleted"
        pos += len(line) + 1


SWEEPS = {f.__name__: f for f in (relational, arith, literal, logic, swap, delete)}


def _run(tmp, name, text):
    d = os.path.join(tmp, name)
    os.makedirs(d)
    src, lib = os.path.join(d, "jslam_oracle.c"), os.path.join(d, "libjslam_oracle.so")
    with open(src, "w") as f:
        f.write(text)
    code = T._DRIVER.format(root=T.ROOT, src=src, lib=lib, pins=T.PINS)
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=60, cwd=T.ROOT)
    except subprocess.TimeoutExpired:
        return "timeout"
    if r.returncode == 1:
        return "caught"
    if r.returncode == 0:
        return "SURVIVED"
    return "does not compile" if "error" in (r.stdout + r.stderr).lower() and r.returncode == 2 else f"rc {r.returncode}"


def main(names):
    for name in names:
        muts = list(SWEEPS[name]())
        print(f"# {name}: {len(muts)} mutants", flush=True)
        with tempfile.TemporaryDirectory() as tmp, ThreadPoolExecutor(max(2, min(8, os.cpu_count() or 2))) as ex:
            futs = [(pos, what, ex.submit(_run, tmp, f"m{k}", text)) for k, (pos, text, what) in enumerate(muts)]
            for pos, what, f in futs:
                verdict = f.result()
                if verdict != "caught":
                    ln, line = _site(pos)
                    print(f"{verdict:16s} line {ln}: {what} | {line}", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(SWEEPS))
